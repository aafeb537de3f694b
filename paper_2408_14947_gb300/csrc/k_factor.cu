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
// memory.  Right-looking Cholesky in panels of kPB = 8 columns; the trailing
// update A22 -= L21 L21^T is a rank-kPB step in TS x TS FP64 register tiles
// over the lower triangle, reading L21 from a column-major copy.  Two panel
// schedules:
//  * column schedule (d <= 128: several CTAs per SM, or one 1024-thread CTA
//    per line when fewer lines than SMs are factored): thread r owns row
//    j0 + r and keeps its panel entries in registers; per column every row
//    scales its entry by 1/l_jj (the panel rows publish theirs), barrier, then
//    updates its later panel entries while the next pivot's row takes
//    l_jj = a_jj rsqrt(a_jj), barrier; then the whole trailing update.  The
//    other resident CTAs fill the FP64 pipe during the barriers;
//  * look-ahead schedule (d > 128, where one CTA fills an SM),
//    three barriers per panel:
//    (1) warp 0 factors the panel's 8 x 8 diagonal block while the other warps
//        apply the previous panel's update to the trailing triangle right of
//        this panel, tiles handed out 32 at a time from a shared counter
//        (warp 0 joins when its block is done);
//    (2) each row below the block computes its panel entries against the block
//        (one thread per row) into A and the L21 copy;
//    (3) the panel's update of the next panel's columns only, so the next
//        block can start at once.
//    The chain of pivots (a reciprocal square root per column) thus runs beside
//    the bulk of the multiply-adds instead of between barriers.
// In both, every element receives the same multiply-adds in the same order as
// in the column-by-column algorithm (a_ik = fma(-l_ij, l_kj, a_ik), j
// ascending), so all variants give the same bits.
// Each diagonal block is then inverted by one warp, one row per lane
// (invert_diag_block, erx_internal.cuh; the FP64 forms: the FP32 routes invert
// them in FP32 in trinv32).  A pivot that is not positive and finite records
// the line in the error slot and poisons its scores (NaN).
#include <cmath>

#include "erx_batch.cuh"
#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kThreads = 256;
constexpr int kNB = kFactorBlock;
constexpr int kPB = 8;             // panel width
// smallest d whose lone lines take the cluster factor (below it a line's
// factor is a few microseconds on one SM)
constexpr int kClusterMinD = 48;

__device__ __forceinline__ int pidx(int i, int k) { return i * (i + 1) / 2 + k; }

// rows of the column-major L21 copy (a multiple of 4: whole register tiles of 2 or 4)
__host__ __device__ inline int lp_stride(int d) { return (d + 3) & ~3; }
// shared memory: A (packed, padded to 16 bytes) | L21 copy [kPB][lp_stride] | 1/l_jj [d]
__host__ __device__ inline size_t chol_smem(int d) {
  return (size_t)(((packed_size(d) + 1) & ~1) + kPB * lp_stride(d) + d) * sizeof(double);
}

// Factor one line's K (packed, src) into the blocked factor (dst, dst32);
// `line` is the global line index reported on a bad pivot.  TS: edge of the
// trailing update's register tiles (2 x 2 everywhere: 4 x 4 tiles need fewer
// shared-memory loads per DFMA, but their 8k-cycle chunks leave a long uneven
// tail at every barrier; measured 12 % slower at d = 224).  LA: the look-ahead
// schedule (d > 128, one CTA per SM, where barriers cannot be hidden by other
// CTAs); else the column schedule (several CTAs per SM, where the look-ahead's
// one-warp block factor costs more FP64 issue slots than the barriers it
// saves, and single lines at d <= 128, where its block chain is the longer).
template <int TS, int NT = kThreads, bool LA = false>
__device__ __forceinline__ void chol_body(const double* __restrict__ src, int d, double ridge,
                                          double* __restrict__ dst, float* __restrict__ d32,
                                          unsigned long long* __restrict__ err, int64_t line,
                                          bool inv) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double Pl[kPB][kPB];   // Pl[r][c] = l_{j0+r, j0+c}: the panel rows' scaled entries
  __shared__ double s_ri[kPB];      // 1 / l_jj of the panel's columns
  __shared__ int s_next;            // next trailing tile to hand out (look-ahead)
  const int P = d * (d + 1) / 2;
  const int ls = lp_stride(d);
  double* A = sm;
  double* Lp = sm + ((P + 1) & ~1);
  double* rdiag = Lp + kPB * ls;    // 1 / l_jj
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int q = tid; q < P; q += NT) A[q] = src[q];
  if (tid == 0) s_next = 0;
  __syncthreads();
  for (int j = tid; j < d; j += NT) A[pidx(j, j)] += ridge;
  __syncthreads();

  // rank-jbp update of the TS x TS tile (I, J) of the lower triangle whose tile
  // grid starts at row and column g; Lp row r holds l_{g+r, c} of the panel
  auto tile = [&](int g, int I, int J, int jbp) {
    double acc[TS][TS];
#pragma unroll
    for (int u = 0; u < TS; ++u)
#pragma unroll
      for (int v = 0; v < TS; ++v) {
        const int gi = g + TS * I + u, gk = g + TS * J + v;
        acc[u][v] = (gi < d && gk <= gi) ? A[pidx(gi, gk)] : 0.0;
      }
    constexpr int kU = TS == 4 ? 2 : kPB;   // 4 x 4 tiles: no room to hoist more loads
#pragma unroll kU
    for (int c = 0; c < jbp; ++c) {
      double av[TS], bv[TS];
#pragma unroll
      for (int h = 0; h < TS; h += 2) {
        const double2 x = *reinterpret_cast<const double2*>(Lp + c * ls + TS * I + h);
        const double2 y = *reinterpret_cast<const double2*>(Lp + c * ls + TS * J + h);
        av[h] = x.x, av[h + 1] = x.y, bv[h] = y.x, bv[h + 1] = y.y;
      }
#pragma unroll
      for (int u = 0; u < TS; ++u)
#pragma unroll
        for (int v = 0; v < TS; ++v) acc[u][v] = fma(-av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < TS; ++u)
#pragma unroll
      for (int v = 0; v < TS; ++v) {
        const int gi = g + TS * I + u, gk = g + TS * J + v;
        if (gi < d && gk <= gi) A[pidx(gi, gk)] = acc[u][v];
      }
  };
  // tile q of a triangle of tiles -> (I, J), J <= I
  auto tri = [](int q, int& I, int& J) {
    I = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
    while (I * (I + 1) / 2 > q) --I;
    while ((I + 1) * (I + 2) / 2 <= q) ++I;
    J = q - I * (I + 1) / 2;
  };
  // pivot of column j (its updated diagonal a): l_jj = a rsqrt(a), published
  auto pivot = [&](double& a, int jj, int j) {
    if (!(a > 0.0) || !isfinite(a)) {
      atomicMin(&err[kErrNotPD], (unsigned long long)line);
      a = __longlong_as_double(0x7ff8000000000000ll);
    }
    const double ri = rsqrt(a);
    s_ri[jj] = ri;
    rdiag[j] = ri;
    a = a * ri;
  };

  if constexpr (LA) {
    constexpr int J0 = kPB / TS;      // tile columns of one panel
    static_assert(NT >= kMaxDim, "step (2) takes one row per thread");
    for (int j0 = 0; j0 < d; j0 += kPB) {
      const int jb = min(kPB, d - j0);
      // (1) warp 0 factors the panel's diagonal block in Pl (lane r owns row r)
      //     while the other warps, and warp 0 once done, apply the previous
      //     panel's update to the columns right of this panel
      if (warp == 0) {
        const int r = lane;
        if (r < jb)
          for (int c = 0; c <= r; ++c) Pl[r][c] = A[pidx(j0 + r, j0 + c)];
        __syncwarp();
        for (int jj = 0; jj < jb; ++jj) {
          if (r == jj) pivot(Pl[jj][jj], jj, j0 + jj);
          __syncwarp();
          if (r > jj && r < jb) Pl[r][jj] = Pl[r][jj] * s_ri[jj];
          __syncwarp();
          if (r > jj && r < jb) {
            const double l = Pl[r][jj];
            for (int c = jj + 1; c <= r; ++c) Pl[r][c] = fma(-l, Pl[c][jj], Pl[r][c]);
          }
          __syncwarp();
        }
        if (r < jb)
          for (int c = 0; c <= r; ++c) A[pidx(j0 + r, j0 + c)] = Pl[r][c];
      }
      if (j0 > 0) {
        const int nt = (d - j0 + TS - 1) / TS, n2 = nt - J0;
        const int ntile = n2 > 0 ? n2 * (n2 + 1) / 2 : 0;
        for (;;) {
          int base = 0;
          if (lane == 0) base = atomicAdd(&s_next, 32);
          base = __shfl_sync(0xffffffffu, base, 0);
          if (base >= ntile) break;
          const int q = base + lane;
          if (q < ntile) {
            int I, J;
            tri(q, I, J);
            tile(j0, I + J0, J + J0, kPB);
          }
        }
      }
      __syncthreads();
      // (2) the rows below the block: their panel entries against the block,
      //     into A and the column-major copy (zero rows pad whole tiles)
      const int g = j0 + jb, m = d - g;
      const int mr = ((m + TS - 1) / TS) * TS;
      if (tid == 0) s_next = 0;
      if (const int t = tid; t < mr) {
        const int i = g + t;
        double a[kPB];
#pragma unroll
        for (int c = 0; c < kPB; ++c) a[c] = (t < m && c < jb) ? A[pidx(i, j0 + c)] : 0.0;
        if (t < m) {
#pragma unroll
          for (int c = 0; c < kPB; ++c) {
            if (c >= jb) break;
            const double l = a[c] * s_ri[c];
            a[c] = l;
#pragma unroll
            for (int c2 = c + 1; c2 < kPB; ++c2)
              if (c2 < jb) a[c2] = fma(-l, Pl[c2][c], a[c2]);
          }
#pragma unroll
          for (int c = 0; c < kPB; ++c)
            if (c < jb) A[pidx(i, j0 + c)] = a[c];
        }
#pragma unroll
        for (int c = 0; c < kPB; ++c) Lp[c * ls + t] = a[c];
      }
      __syncthreads();
      // (3) this panel's update of the next panel's columns (rows >= g)
      if (m > 0) {
        const int nt = mr / TS, jn = min(J0, nt);
        const int ntile = jn * nt - jn * (jn - 1) / 2;   // sum over J < jn of (nt - J)
        for (int q = tid; q < ntile; q += NT) {
          int J = 0, rem = q;
          while (rem >= nt - J) rem -= nt - J, ++J;
          tile(g, J + rem, J, jb);
        }
      }
      __syncthreads();
    }
  } else {
    for (int j0 = 0; j0 < d; j0 += kPB) {
      const int jb = min(kPB, d - j0);
      const int rl = tid, i = j0 + rl;          // this thread's row (d - j0 <= NT)
      const bool own = i < d;
      double a[kPB];
#pragma unroll
      for (int c = 0; c < kPB; ++c) a[c] = (own && c < jb && c <= rl) ? A[pidx(i, j0 + c)] : 0.0;
      if (own && rl == 0) pivot(a[0], 0, j0);
      __syncthreads();
#pragma unroll
      for (int jj = 0; jj < kPB; ++jj) {
        if (jj >= jb) break;
        // scale this row's entry of column jj; panel rows publish theirs
        double lij = 0.0;
        if (own && rl > jj) {
          lij = a[jj] * s_ri[jj];
          a[jj] = lij;
          if (rl < jb) Pl[rl][jj] = lij;
        }
        __syncthreads();
        // update this row's later panel entries; the next pivot's row takes its pivot
        if (own && rl > jj) {
#pragma unroll
          for (int c = jj + 1; c < kPB; ++c)
            if (c < jb && c <= rl) a[c] = fma(-lij, Pl[c][jj], a[c]);
          if (rl == jj + 1 && rl < jb) pivot(a[min(jj + 1, kPB - 1)], jj + 1, i);
        }
        __syncthreads();
      }
      // the panel's final entries back into A; L21 (rows below the panel) into
      // its column-major copy, zero-padded to whole tiles
      if (own) {
#pragma unroll
        for (int c = 0; c < kPB; ++c)
          if (c < jb && c <= rl) A[pidx(i, j0 + c)] = a[c];
      }
      const int m = d - j0 - jb;                 // trailing rows
      const int r2 = rl - jb;
      if (r2 >= 0 && r2 < ((m + TS - 1) / TS) * TS) {
#pragma unroll
        for (int c = 0; c < kPB; ++c) Lp[c * ls + r2] = (r2 < m && c < jb) ? a[c] : 0.0;
      }
      __syncthreads();
      if (m > 0) {
        const int nt = (m + TS - 1) / TS;
        const int ntile = nt * (nt + 1) / 2;
        for (int q = tid; q < ntile; q += NT) {
          int I, J;
          tri(q, I, J);
          tile(j0 + jb, I, J, jb);
        }
      }
      __syncthreads();
    }
  }

  __syncthreads();
  // invert each 32 x 32 diagonal block in place, warp w taking blocks w, w + 8, ...
  const int nblk = inv ? (d + kNB - 1) / kNB : 0;
  for (int bk = warp; bk < nblk; bk += NT / 32)
    invert_diag_block<1>(A, bk * kNB, min(kNB, d - bk * kNB), rdiag + bk * kNB, 0, lane);
  __syncthreads();
  for (int q = threadIdx.x; q < P; q += NT) dst[q] = A[q];
  if (d32) {
    for (int q = threadIdx.x; q < P; q += NT) d32[q] = (float)A[q];
  }
}

template <int TS, int MINB, int NT = kThreads, bool LA = false>
__global__ void __launch_bounds__(NT, MINB) chol_kernel(const double* __restrict__ K_t, int d,
                                                    double ridge, double* __restrict__ Lf,
                                                    float* __restrict__ Lf32,
                                                    unsigned long long* __restrict__ err,
                                                    int64_t t0, bool inv) {
  const int t = blockIdx.x;
  const int64_t P = packed_size(d);
  chol_body<TS, NT, LA>(K_t + t * P, d, ridge, Lf + t * P, Lf32 ? Lf32 + t * P : nullptr, err,
                    t0 + t, inv);
}

// Batched form: one CTA per stream, streams taken from a work list (largest d
// first).  NT / LA as for the single-stream kernel: d > 128 takes the
// look-ahead schedule with 512 threads (one CTA per SM), the others the column
// schedule with 256 threads (several CTAs per SM).  A bad pivot records the
// stream index.
template <int NT, bool LA>
__global__ void __launch_bounds__(NT, LA ? 1 : 4) b_chol_kernel(const BStream* __restrict__ S,
                                                               const BItem* __restrict__ items,
                                                               bool want32,
                                                               unsigned long long* __restrict__ err) {
  const int si = items[blockIdx.x].s;
  const BStream& s = S[si];
  // the FP32 routes invert the diagonal blocks in trinv32 (FP32)
  chol_body<2, NT, LA>(s.K_t, s.d, s.ridge, s.Lf, want32 ? s.Lf32 : nullptr, err, si, !want32);
}

// Full inverse X = L^{-1} in FP32 from the float factor (plain diagonal blocks:
// the FP32 routes skip the FP64 block inversion), for the FP32, TF32, BF16 and
// 3xTF32 forms (their score kernels then apply X with one triangular
// product instead of a block-by-block solve).  One CTA per line, in place in
// shared memory and in the caller's buffer.  Column blocks left to right, row
// blocks top to bottom:  X_KK = D_K (already stored),
//   X_JK = -D_J (sum_{M=K}^{J-1} L_JM X_MK),   J > K,
// which reads only L entries of rows >= J and X entries of column block K
// above row block J, so X_JK can overwrite L_JK.  d^3/6 FP32 multiply-adds.
__device__ __forceinline__ void trinv32_body(float* __restrict__ Lf32, int d) {
  static_assert(kThreads == 256 && kNB == 32, "one 2 x 2 tile per thread covers a 32 x 32 block");
  extern __shared__ __align__(16) float S[];
  __shared__ float Tm[kNB * kNB];
  const int P = d * (d + 1) / 2;
  for (int q = threadIdx.x; q < P; q += kThreads) S[q] = Lf32[q];
  __syncthreads();
  const int nblk = (d + kNB - 1) / kNB;
  // the factor comes with plain diagonal blocks L_KK: D_K = L_KK^{-1} first, in
  // FP32, one warp per block, columns right to left (column j becomes
  // -(1/l_jj) T l_col with T the already inverted trailing part; lane i: row i)
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bk = warp; bk < nblk; bk += kThreads / 32) {
      const int j0 = bk * kNB, nb = min(kNB, d - j0);
      for (int j = nb - 1; j >= 0; --j) {
        const float rjj = 1.0f / S[pidx(j0 + j, j0 + j)];
        const int i = lane;
        float acc = 0.f;
        if (i > j && i < nb) {
          const float* Ti = S + pidx(j0 + i, j0);
          for (int k = j + 1; k <= i; ++k) acc = fmaf(Ti[k], S[pidx(j0 + k, j0 + j)], acc);
        }
        __syncwarp();
        if (i > j && i < nb) S[pidx(j0 + i, j0 + j)] = -rjj * acc;
        if (i == j) S[pidx(j0 + j, j0 + j)] = rjj;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  for (int K = 0; K < nblk; ++K) {
    const int k0 = K * kNB, k1 = min(d, k0 + kNB);
    for (int J = K + 1; J < nblk; ++J) {
      const int j0 = J * kNB, j1 = min(d, j0 + kNB);
      // each thread a 2 x 2 tile: rows j, j+1 and columns k, k+1 of the pair
      // (kThreads = 256 tiles = 32 x 32 entries); every entry keeps its own
      // chain of multiply-adds in the order of the one-entry loop
      const int jj = 2 * (threadIdx.x >> 4), kk = 2 * (threadIdx.x & 15);
      const int j = j0 + jj, k = k0 + kk;
      const bool vj = j < j1, vj1 = j + 1 < j1, vk = k < k1, vk1 = k + 1 < k1;
      // T = sum_M L_JM X_MK over columns m in [k0, j0)
      {
        float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
        if (vj && vk) {
          const float* L0 = S + pidx(j, 0);
          const float* L1 = vj1 ? S + pidx(j + 1, 0) : L0;
          // m = k: column k only (X_{k, k+1} lies above the diagonal)
          const float xkk = S[pidx(k, k)];
          a00 = fmaf(L0[k], xkk, a00);
          a10 = fmaf(L1[k], xkk, a10);
          for (int m = k + 1; m < j0; ++m) {
            const float* Xm = S + pidx(m, k);      // X_mk, X_m,k+1 (k + 1 <= m)
            const float x0 = Xm[0], x1 = Xm[1], l0 = L0[m], l1 = L1[m];
            a00 = fmaf(l0, x0, a00);
            a01 = fmaf(l0, x1, a01);
            a10 = fmaf(l1, x0, a10);
            a11 = fmaf(l1, x1, a11);
          }
        }
        Tm[jj * kNB + kk] = a00;
        Tm[jj * kNB + kk + 1] = a01;
        Tm[(jj + 1) * kNB + kk] = a10;
        Tm[(jj + 1) * kNB + kk + 1] = a11;
      }
      __syncthreads();
      // X_JK = -D_J T (D_J lower triangular, rows j, cols i <= j of block J)
      if (vj && vk) {
        const float* D0 = S + pidx(j, j0);
        const float* D1 = vj1 ? S + pidx(j + 1, j0) : D0;
        float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
        for (int ii = 0; ii <= jj; ++ii) {
          const float t0 = Tm[ii * kNB + kk], t1 = Tm[ii * kNB + kk + 1];
          const float d0 = D0[ii], d1 = D1[ii];
          a00 = fmaf(d0, t0, a00);
          a01 = fmaf(d0, t1, a01);
          a10 = fmaf(d1, t0, a10);
          a11 = fmaf(d1, t1, a11);
        }
        if (vj1) {   // row j+1 has one more term, its diagonal
          const float d1 = D1[jj + 1];
          a10 = fmaf(d1, Tm[(jj + 1) * kNB + kk], a10);
          a11 = fmaf(d1, Tm[(jj + 1) * kNB + kk + 1], a11);
        }
        S[pidx(j, k)] = -a00;
        if (vk1) S[pidx(j, k + 1)] = -a01;
        if (vj1) S[pidx(j + 1, k)] = -a10;
        if (vj1 && vk1) S[pidx(j + 1, k + 1)] = -a11;
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < P; q += kThreads) Lf32[q] = S[q];
}

__global__ void __launch_bounds__(kThreads) trinv32_kernel(float* __restrict__ Lf32, int d) {
  trinv32_body(Lf32 + (int64_t)blockIdx.x * packed_size(d), d);
}

__global__ void __launch_bounds__(kThreads) b_trinv32_kernel(const BStream* __restrict__ S,
                                                             const BItem* __restrict__ items) {
  const BStream& s = S[items[blockIdx.x].s];
  trinv32_body(s.Lf32, s.d);
}

}  // namespace

void launch_trinv32(float* Lf32, int d, int T, cudaStream_t st) {
  trinv32_kernel<<<T, kThreads, (size_t)packed_size(d) * sizeof(float), st>>>(Lf32, d);
}

void launch_batch_trinv32(const BStream* S, const BItem* items, int n, int dmax,
                          cudaStream_t st) {
  if (n > 0)
    b_trinv32_kernel<<<n, kThreads, (size_t)packed_size(dmax) * sizeof(float), st>>>(S, items);
}

// clusters of the cluster factor that fit on the device at once (0: not used)
int& cluster_slots() {
  static int n = 0;
  return n;
}

cudaError_t configure_factor_kernels() {
  const int m = (int)chol_smem(kMaxDim);
  cudaError_t e =
      cudaFuncSetAttribute(chol_kernel<2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_kernel<2, 1, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_kernel<2, 1, 512, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(b_chol_kernel<kThreads, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(b_chol_kernel<512, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, m);
  if (e == cudaSuccess) cluster_slots() = configure_cluster_factor(device_shape().smem_per_sm);
  const int m32 = (int)(packed_size(kMaxDim) * sizeof(float));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(trinv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m32);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(b_trinv32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, m32);
  return e;
}

void launch_batch_chol(const BStream* S, const BItem* items, int n, int dmax, bool big,
                       bool want32, unsigned long long* err, cudaStream_t st) {
  if (n <= 0) return;
  if (big)
    b_chol_kernel<512, true><<<n, 512, chol_smem(dmax), st>>>(S, items, want32, err);
  else
    b_chol_kernel<kThreads, false><<<n, kThreads, chol_smem(dmax), st>>>(S, items, want32, err);
}

void launch_chol_inv(const double* K_t, int d, int T, double ridge, double* Lf, float* Lf32,
                     unsigned long long* err, int64_t t0, cudaStream_t st, bool invert,
                     bool leave_room) {
  // above 128 dimensions the factor fills an SM's shared memory: one CTA per SM.
  // Fewer lines than SMs (a line or a few pushed alone): one CTA per SM anyway,
  // so each takes more threads (as many as its registers allow) to hide the
  // latency of its barriers and DFMA chains.
  const int n_sm = device_shape().n_sm, smem_sm = device_shape().smem_per_sm;
  const size_t sm = chol_smem(d);
  // d > 128: one CTA per SM, look-ahead schedule.  Fewer lines than SMs at
  // d <= 128 (a line pushed alone): the column schedule with 1024 threads, whose
  // pivot chain is shorter than the look-ahead's one-warp block chain there
  // (measured: 27 us more per line with the look-ahead at d = 108).
  // A line or a few pushed alone at d >= kClusterMinD: each over a cluster of
  // SMs (k_factor_cluster.cu), as long as all clusters are resident at once.
  if (d >= kClusterMinD && T <= cluster_slots() && T * chol_cluster_ctas() <= n_sm)
    launch_chol_cluster(K_t, d, T, ridge, Lf, Lf32, err, t0, invert, smem_sm, st);
  else if (d > 128)
    chol_kernel<2, 1, 512, true><<<T, 512, sm, st>>>(K_t, d, ridge, Lf, Lf32, err, t0, invert);
  else if (T < n_sm)
    chol_kernel<2, 1, 1024><<<T, 1024, sm, st>>>(K_t, d, ridge, Lf, Lf32, err, t0, invert);
  else {
    // leave_room: at most three CTAs per SM (a quarter of the SM's shared memory
    // requested), so the score kernels of the previous block, on another
    // stream, find registers and shared memory beside the factor
    const size_t room = smem_sm > 0 ? (size_t)smem_sm / 4 + 1024 : sm;
    const size_t smr = leave_room && room > sm ? room : sm;
    chol_kernel<2, 4><<<T, kThreads, smr, st>>>(K_t, d, ridge, Lf, Lf32, err, t0, invert);
  }
}

}  // namespace erx

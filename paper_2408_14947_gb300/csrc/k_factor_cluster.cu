// S4 (Sec. III-D) for a line, or a few, pushed alone: one line's factor
// L_t = chol(K_t + ridge I) over a cluster of kCl CTAs, with the arithmetic of
// the one-CTA kernels of k_factor.cu, so the blocked factor it writes is bit
// for bit theirs.
//
// On GB300 a warp's DFMA holds the SM's FP64 pipe for ~19 cycles and a
// dependent DFMA waits 64, so one line's d^3/6 multiply-adds at d = 108 keep
// a single SM busy for ~60 us on their own, and the pivot chain (a double
// reciprocal square root, ~370 cycles, per column) adds to that.  Here the
// work is split by role:
//  * CTA 0, the master, runs the chain that cannot be spread: it factors
//    column panel p (kPB = 8 columns; pivots, scaling and the panel's own
//    updates, one thread per row, exactly as the column schedule), writes the
//    panel's final entries, publishes its L below the panel in a ring slot of
//    its shared memory, applies panel p to panel p + 1 and goes on with p + 1;
//  * the helpers (CTAs 1 .. kCl - 1) own the panels q >= 2, dealt out
//    cyclically, and keep them current: for each published panel p they copy
//    its L through distributed shared memory and apply it to their panels
//    q >= p + 2, panel p + 2 first, which then goes to the master (current
//    through panel p) into the buffer the master has just finished with.
//    The trailing update, the bulk of the multiply-adds, thus runs on the
//    helpers' FP64 pipes beside the master's chain;
//  * each 32 x 32 diagonal block is inverted by a helper as soon as its last
//    panel is final (FP64 forms).
// Every entry receives the same multiply-adds in the same order as in the
// column-by-column algorithm (panel by panel, j ascending), and the pivots and
// the inversion are the same code, hence the same bits.
// Flags live in shared memory and are read with acquire / written with
// release at cluster scope.  Every wait is bounded: a wait that runs out
// records kErrTimeout, tells every CTA of the cluster to stop, and all CTAs
// meet at the final cluster barrier (no CTA leaves while another may still
// read its shared memory).
#include <cmath>

#include "erx_internal.cuh"

namespace erx {
namespace {

constexpr int kCl = 8;                               // CTAs per line
constexpr int kH = kCl - 1;                          // helpers
constexpr int kNT = 256;                             // threads per CTA (one row each on the master)
constexpr int kPB = 8;                               // panel width
constexpr int kRing = 3;                             // published panels in flight
constexpr int kLs = (kMaxDim + 3) & ~3;              // rows of a column-major panel copy
constexpr int kMaxPan = (kMaxDim + kPB - 1) / kPB;   // 28 panels at most
constexpr int kMaxOwn = (kMaxPan - 2 + kH - 1) / kH; // panels per helper
constexpr int kPanel = kMaxDim * kPB;                // doubles of a row-major panel
constexpr int kNB = kFactorBlock;
constexpr int kBlkP = kNB * (kNB + 1) / 2;           // a packed diagonal block
constexpr unsigned kWaitLimit = 1u << 22;            // polls before a wait gives up
static_assert(kNT >= kMaxDim, "the master takes one row per thread");

// dynamic shared memory, in doubles (the same layout offsets in every CTA)
//   master: CP[2] (panels p, p + 1; row-major [row][kPB]) | LB[kRing] ([kPB][kLs]) | RD[kMaxDim]
//   helper: OWN[kMaxOwn] (row-major panels) | LH ([kPB][kLs]) | IB (packed block) | IR[kNB]
constexpr int kOffCP = 0, kOffLB = 2 * kPanel, kOffRD = kOffLB + kRing * kPB * kLs;
constexpr int kOffOwn = 0, kOffLH = kMaxOwn * kPanel, kOffIB = kOffLH + kPB * kLs,
              kOffIR = kOffIB + kBlkP;
constexpr int kSmemDoubles = (kOffRD + kMaxDim) > (kOffIR + kNB) ? (kOffRD + kMaxDim)
                                                                  : (kOffIR + kNB);

__device__ __forceinline__ int pidx(int i, int k) { return i * (i + 1) / 2 + k; }

// ---- cluster primitives ---------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t remote(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned ld_acquire(uint32_t a) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t a, unsigned v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void add_release(uint32_t a, unsigned v) {
  asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v)
               : "memory");
}
__device__ __forceinline__ double2 ld_remote2(uint32_t a) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ double ld_remote(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void st_remote2(uint32_t a, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y)
               : "memory");
}
__device__ __forceinline__ void fence_cluster() {
  asm volatile("fence.acq_rel.cluster;" ::: "memory");
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

struct Flags {
  unsigned pub;            // master: panels published
  unsigned cp[2];          // master: q + 1 of the panel delivered into CP[q & 1]
  unsigned used[kRing];    // master: helper copies taken of ring slot s
  unsigned blk;            // master: diagonal blocks whose entries are in memory
  unsigned stop;           // every CTA: nonzero once any wait of the cluster ran out
  int ok;                  // CTA-wide result of the last wait
};

// Thread 0: wait until the flag at shared::cluster address a is >= v.  Gives up when
// the cluster is told to stop or after kWaitLimit polls; then records the line
// in the timeout slot and tells every CTA to stop.
__device__ bool wait_ge(Flags& f, uint32_t a, unsigned v, unsigned long long* err,
                        int64_t line) {
  const uint32_t stop = remote(saddr(&f.stop), cta_rank());
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    if (ld_acquire(a) >= v) return true;
    if (ld_acquire(stop) != 0u) return false;
  }
  atomicMin(&err[kErrTimeout], (unsigned long long)line);
  for (uint32_t r = 0; r < (uint32_t)kCl; ++r) st_release(remote(saddr(&f.stop), r), 1u);
  return false;
}
// the whole CTA waits on thread 0's wait; returns the shared verdict
__device__ __forceinline__ bool cta_wait(Flags& f, uint32_t a, unsigned v,
                                         unsigned long long* err, int64_t line) {
  __syncthreads();   // every thread has read the previous verdict
  if (threadIdx.x == 0) f.ok = wait_ge(f, a, v, err, line) ? 1 : 0;
  __syncthreads();
  const bool ok = f.ok != 0;
  if (ok) fence_cluster();
  return ok;
}

// ---- panels -----------------------------------------------------------------
// Panel q of K + ridge I (rows 8q .. d-1, its columns; row-major [row][kPB],
// entries above the diagonal and beyond the panel zero).
__device__ void load_panel(double* __restrict__ C, const double* __restrict__ K, int d, int q,
                           double ridge) {
  const int q0 = q * kPB, jb = min(kPB, d - q0), n = (d - q0) * kPB;
  // eight loads in flight per thread before their stores
  for (int e0 = threadIdx.x; e0 < n; e0 += 8 * kNT) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kNT, r = e / kPB, c = e - r * kPB;
      v[u] = (e < n && c < jb && c <= r) ? __ldg(K + pidx(q0 + r, q0 + c)) : 0.0;
      if (e < n && c == r && c < jb) v[u] += ridge;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u * kNT < n) C[e0 + u * kNT] = v[u];
  }
}

// Apply panel p's rank-jbp update to panel C (first row and column q0, jbq
// columns): a_ic = fma(-l_ij, l_cj, a_ic) for j ascending, i >= c.  L of panel
// p below it is column-major in Lp (row x at Lp[j * kLs + x - g], rows from g,
// zero-padded to an even count).  2 x 2 tiles of (row, column) pairs.
__device__ void apply_panel(double* __restrict__ C, int q0, int jbq, int d,
                            const double* __restrict__ Lp, int g, int jbp) {
  const int nr = d - q0;
  const int tu = (nr + 1) >> 1, tv = (jbq + 1) >> 1;
  for (int t = threadIdx.x; t < tu * tv; t += kNT) {
    const int U = t / tv, V = t - U * tv;
    if (2 * V > 2 * U + 1) continue;            // wholly above the diagonal
    double acc[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int r = 2 * U + u, c = 2 * V + v;
        acc[u][v] = (r < nr && c < jbq && c <= r) ? C[r * kPB + c] : 0.0;
      }
    const double* Li = Lp + (q0 + 2 * U - g);
    const double* Lc = Lp + (q0 + 2 * V - g);
#pragma unroll
    for (int j = 0; j < kPB; ++j) {
      if (j >= jbp) break;
      const double2 a = *reinterpret_cast<const double2*>(Li + j * kLs);
      const double2 b = *reinterpret_cast<const double2*>(Lc + j * kLs);
      acc[0][0] = fma(-a.x, b.x, acc[0][0]);
      acc[0][1] = fma(-a.x, b.y, acc[0][1]);
      acc[1][0] = fma(-a.y, b.x, acc[1][0]);
      acc[1][1] = fma(-a.y, b.y, acc[1][1]);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int r = 2 * U + u, c = 2 * V + v;
        if (r < nr && c < jbq && c <= r) C[r * kPB + c] = acc[u][v];
      }
  }
}

// the master's rows: row blocks 0-5 (32 rows each) on warps 1, 2, 3, 5, 6, 7 and
// block 6 on warp 4, so that warp 0 and its SM sub-partition stay free for the
// pivots (warp 4, on the same sub-partition, takes rows only beyond 192)
static_assert(7 * 32 >= kMaxDim, "seven row warps cover the largest panel");
__device__ __forceinline__ int row_of_thread(int tid) {
  const int w = tid >> 5, lane = tid & 31;
  const int k = w == 0 ? -1 : w < 4 ? w - 1 : w == 4 ? 6 : w - 2;
  return k < 0 ? -1 : 32 * k + lane;
}

// the helper that owns panel q >= 2
__device__ __forceinline__ int owner_of(int q) { return 1 + (q - 2) % kH; }
// the last panel of diagonal block b, and the helper that inverts it: the one
// whose next panel due at the master is furthest off (it sent panel lp + 2 - kH
// + ... long ago and owes lp + 4 two panels later)
__device__ __forceinline__ int last_panel(int b, int np) { return min(np - 1, 4 * b + 3); }
__device__ __forceinline__ int inverter_of(int b, int np) { return owner_of(last_panel(b, np) + 4); }

// ---- master: the panel chain ---------------------------------------------------
__device__ void master(Flags& f, double* __restrict__ sm, const double* __restrict__ K, int d,
                       double ridge, double* __restrict__ dst, float* __restrict__ d32, bool inv,
                       unsigned long long* __restrict__ err, int64_t line) {
  __shared__ double Pl[kPB][kPB];   // Pl[r][c] = l_{j0+r, j0+c}: the panel rows' scaled entries
  __shared__ double s_ri[kPB];      // 1 / l_jj of the panel's columns
  __shared__ double s_piv[2];       // the next pivot's updated diagonal, and its l_jj
  double* CP = sm + kOffCP;
  double* LB = sm + kOffLB;
  double* RD = sm + kOffRD;
  const int tid = threadIdx.x;
  const int np = (d + kPB - 1) / kPB;
  auto pivot = [&](double& a, int jj, int j) {
    if (!(a > 0.0) || !isfinite(a)) {
      atomicMin(&err[kErrNotPD], (unsigned long long)line);
      a = __longlong_as_double(0x7ff8000000000000ll);
    }
    const double ri = rsqrt(a);
    s_ri[jj] = ri;
    RD[j] = ri;
    a = a * ri;
  };
  load_panel(CP, K, d, 0, ridge);
  if (np > 1) load_panel(CP + kPanel, K, d, 1, ridge);
  __syncthreads();
  for (int p = 0; p < np; ++p) {
    const int j0 = p * kPB, jb = min(kPB, d - j0), m = d - j0;
    const double* C = CP + (p & 1) * kPanel;
    // (1) the column schedule of k_factor.cu on this panel.  Row rl of the panel
    //     is on the thread row_of_thread maps to it; thread 0 (warp 0) takes the
    //     pivots, alone on its SM sub-partition's FP64 unit while the panel has at
    //     most 192 rows.  Per column the next pivot's row scales its entry and
    //     updates its diagonal first and hands it over; the pivot then runs while
    //     the other rows update their entries on the other sub-partitions.
    //     Every entry gets the same operations as in the one-CTA kernels.
    const int rl = row_of_thread(tid), i = j0 + rl;
    const bool own = rl >= 0 && rl < m;
    double a[kPB];
#pragma unroll
    for (int c = 0; c < kPB; ++c) a[c] = (own && c < jb && c <= rl) ? C[rl * kPB + c] : 0.0;
    if (own && rl == 0) s_piv[0] = a[0];
    __syncthreads();
    if (tid == 0) {
      double v = s_piv[0];
      pivot(v, 0, j0);
      s_piv[1] = v;
    }
    __syncthreads();
    if (own && rl == 0) a[0] = s_piv[1];
#pragma unroll
    for (int jj = 0; jj < kPB; ++jj) {
      if (jj >= jb) break;
      const int jn = min(jj + 1, kPB - 1);
      const bool nxt = own && rl == jj + 1 && rl < jb;   // the next pivot's row
      double lij = 0.0;
      if (own && rl > jj) {
        lij = a[jj] * s_ri[jj];
        a[jj] = lij;
        if (rl < jb) Pl[rl][jj] = lij;
        if (nxt) {
          a[jn] = fma(-lij, lij, a[jn]);   // its own entry of column jj: Pl[jj + 1][jj] = lij
          s_piv[0] = a[jn];
        }
      }
      __syncthreads();
      if (tid == 0 && jj + 1 < jb) {
        double v = s_piv[0];
        pivot(v, jj + 1, j0 + jj + 1);
        s_piv[1] = v;
      }
      if (own && rl > jj) {
#pragma unroll
        for (int c = jj + 1; c < kPB; ++c)
          if (c < jb && c <= rl && !(nxt && c == jj + 1)) a[c] = fma(-lij, Pl[c][jj], a[c]);
      }
      __syncthreads();
      if (nxt) a[jn] = s_piv[1];
    }
    // (2) the panel's L below it into ring slot p % kRing, once the helpers have
    //     all copied the panel that used the slot before; then its final entries
    const int s = p % kRing;
    if (p >= kRing &&
        !cta_wait(f, remote(saddr(&f.used[s]), 0), (unsigned)(kH * (p / kRing)), err, line))
      break;
    double* Lb = LB + s * (kPB * kLs);
    const int mb = m - jb, mr = (mb + 1) & ~1;
    const int r2 = rl - jb;
    if (r2 >= 0 && r2 < mr) {
#pragma unroll
      for (int c = 0; c < kPB; ++c) Lb[c * kLs + r2] = (r2 < mb && c < jb) ? a[c] : 0.0;
    }
    fence_cluster();             // 1/l_jj and the slot before the flag
    __syncthreads();
    if (tid == 0) st_release(remote(saddr(&f.pub), 0), (unsigned)(p + 1));
    if (own) {
#pragma unroll
      for (int c = 0; c < kPB; ++c)
        if (c < jb && c <= rl) {
          dst[pidx(i, j0 + c)] = a[c];
          if (d32) d32[pidx(i, j0 + c)] = (float)a[c];
        }
    }
    // the last panel of a diagonal block: its entries are in memory before its
    // inverter reads them
    if (inv && (p == np - 1 || (p & 3) == 3)) {
      fence_cluster();
      __syncthreads();
      if (tid == 0) st_release(remote(saddr(&f.blk), 0), (unsigned)(p / 4 + 1));
    }
    // (3) panel p + 1 (from its helper, current through panel p - 1) gets panel p
    if (p + 1 < np) {
      const int q = p + 1;
      if (q >= 2 && !cta_wait(f, remote(saddr(&f.cp[q & 1]), 0), (unsigned)(q + 1), err, line))
        break;
      apply_panel(CP + (q & 1) * kPanel, q * kPB, min(kPB, d - q * kPB), d, Lb, j0 + jb, jb);
      __syncthreads();
    }
  }
}

// ---- helpers: the trailing panels and the diagonal inverses ---------------------
__device__ void helper(Flags& f, double* __restrict__ sm, int h, const double* __restrict__ K,
                       int d, double ridge, double* __restrict__ dst, float* __restrict__ d32,
                       bool inv, unsigned long long* __restrict__ err, int64_t line) {
  double* OWN = sm + kOffOwn;
  double* LH = sm + kOffLH;
  double* IB = sm + kOffIB;
  double* IR = sm + kOffIR;
  const int tid = threadIdx.x;
  const int np = (d + kPB - 1) / kPB;
  const int nblk = (d + kNB - 1) / kNB;
  // owned panels q = 2 + (h - 1) + k kH, k = 0 .. nown - 1
  const int q_first = 1 + h;
  const int nown = q_first < np ? (np - q_first + kH - 1) / kH : 0;
  const int q_last = q_first + (nown - 1) * kH;
  for (int k = 0; k < nown; ++k) load_panel(OWN + k * kPanel, K, d, q_first + k * kH, ridge);
  __syncthreads();
  const uint32_t pub = remote(saddr(&f.pub), 0);
  for (int p = 0; p < np; ++p) {
    if (!cta_wait(f, pub, (unsigned)(p + 1), err, line)) break;
    const int j0 = p * kPB, jb = min(kPB, d - j0), g = j0 + jb;
    const int mr = (d - g + 1) & ~1;
    const int s = p % kRing;
    if (nown > 0 && q_last >= p + 2) {
      // copy the slot: jb columns of mr rows (pairs of doubles)
      const uint32_t src = remote(saddr(sm + kOffLB + s * (kPB * kLs)), 0);
      const int hr = mr >> 1;
      for (int e = tid; e < jb * hr; e += kNT) {
        const int c = e / hr, r = 2 * (e - c * hr);
        *reinterpret_cast<double2*>(LH + c * kLs + r) =
            ld_remote2(src + (uint32_t)(c * kLs + r) * 8u);
      }
    }
    __syncthreads();
    if (tid == 0) add_release(remote(saddr(&f.used[s]), 0), 1u);
    for (int k = 0; k < nown; ++k) {
      const int q = q_first + k * kH;
      if (q < p + 2) continue;
      double* C = OWN + k * kPanel;
      apply_panel(C, q * kPB, min(kPB, d - q * kPB), d, LH, g, jb);
      __syncthreads();
      if (q == p + 2) {
        // to the master, into the buffer of panel p (done with since it published p)
        const uint32_t dstp = remote(saddr(sm + kOffCP + (q & 1) * kPanel), 0);
        const int n2 = (d - q * kPB) * kPB / 2;
        for (int e = tid; e < n2; e += kNT)
          st_remote2(dstp + (uint32_t)e * 16u, *reinterpret_cast<const double2*>(C + 2 * e));
        fence_cluster();
        __syncthreads();
        if (tid == 0) st_release(remote(saddr(&f.cp[q & 1]), 0), (unsigned)(q + 1));
      }
    }
    // diagonal blocks whose last panel is p and which this helper inverts
    for (int b = 0; inv && b < nblk; ++b) {
      if (last_panel(b, np) != p || inverter_of(b, np) != h) continue;
      const int b0 = b * kNB, nb = min(kNB, d - b0);
      // the block's final L (the master flags it once in memory) and its 1/l_jj
      if (!cta_wait(f, remote(saddr(&f.blk), 0), (unsigned)(b + 1), err, line)) break;
      for (int e = tid; e < kNB * kNB; e += kNT) {
        const int r = e / kNB, c = e - r * kNB;
        if (r < nb && c <= r) IB[pidx(r, c)] = __ldcg(dst + pidx(b0 + r, b0 + c));
      }
      const uint32_t rd = remote(saddr(sm + kOffRD + b0), 0);
      for (int e = tid; e < nb; e += kNT) IR[e] = ld_remote(rd + (uint32_t)e * 8u);
      __syncthreads();
      // four warps, one per SM sub-partition (named barrier 1)
      if (tid < 128) invert_diag_block<4>(IB, 0, nb, IR, tid >> 5, tid & 31, 1);
      __syncthreads();
      for (int e = tid; e < kNB * kNB; e += kNT) {
        const int r = e / kNB, c = e - r * kNB;
        if (r < nb && c <= r) {
          const double v = IB[pidx(r, c)];
          dst[pidx(b0 + r, b0 + c)] = v;
          if (d32) d32[pidx(b0 + r, b0 + c)] = (float)v;
        }
      }
      __syncthreads();
    }
  }
}

// One cluster per line; line t's K at K_t + t P.
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kNT, 1)
    chol_cluster_kernel(const double* __restrict__ K_t, int d, double ridge,
                        double* __restrict__ Lf, float* __restrict__ Lf32,
                        unsigned long long* __restrict__ err, int64_t t0, bool inv) {
  extern __shared__ __align__(16) double sm[];
  __shared__ Flags f;
  const int t = blockIdx.x / kCl;
  const uint32_t rank = cta_rank();
  const int64_t P = packed_size(d);
  if (threadIdx.x == 0) {
    f.pub = 0u;
    f.cp[0] = f.cp[1] = 0u;
    for (int s = 0; s < kRing; ++s) f.used[s] = 0u;
    f.blk = 0u;
    f.stop = 0u;
    f.ok = 1;
  }
  cluster_barrier();   // every CTA's flags are set before any remote access
  const double* K = K_t + t * P;
  double* dst = Lf + t * P;
  float* d32 = Lf32 ? Lf32 + t * P : nullptr;
  if (rank == 0)
    master(f, sm, K, d, ridge, dst, d32, inv, err, t0 + t);
  else
    helper(f, sm, (int)rank, K, d, ridge, dst, d32, inv, err, t0 + t);
  __syncthreads();
  cluster_barrier();   // no CTA leaves while another may read its shared memory
}

}  // namespace

// Shared memory per CTA: the layout above, raised to more than half an SM's
// shared memory so that the cluster's CTAs sit on kCl different SMs (two on
// one SM would share its FP64 pipe).
static size_t chol_cluster_smem(int smem_per_sm) {
  const size_t need = (size_t)kSmemDoubles * sizeof(double);
  const size_t half = smem_per_sm > 0 ? (size_t)smem_per_sm / 2 + 1024 : 0;
  return need > half ? need : half;
}

int configure_cluster_factor(int smem_per_sm) {
  const size_t sm = chol_cluster_smem(smem_per_sm);
  if (cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCl);
  cfg.blockDim = dim3(kNT);
  cfg.dynamicSmemBytes = sm;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = kCl;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, chol_cluster_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int chol_cluster_ctas() { return kCl; }

void launch_chol_cluster(const double* K_t, int d, int T, double ridge, double* Lf, float* Lf32,
                         unsigned long long* err, int64_t t0, bool invert, int smem_per_sm,
                         cudaStream_t st) {
  chol_cluster_kernel<<<T * kCl, kNT, chol_cluster_smem(smem_per_sm), st>>>(
      K_t, d, ridge, Lf, Lf32, err, t0, invert);
}

}  // namespace erx

// GB300 pipe rates and latencies behind the roofline denominators and the
// kernel designs (the derived FP64 peak, the FP64 issue cost of one warp
// instruction, barrier and cluster synchronisation costs).  Built and run by
// `python bench.py --pipe-probe`; prints one JSON object.
//
// Every measurement is a clock64() interval inside one kernel, after a
// warm-up launch; throughputs use all SMs (one resident CTA per SM, several
// independent chains per thread), latencies one thread.  The only waits are
// hardware barriers that every thread reaches and two flag ping-pongs
// between the CTAs of one cluster (co-scheduled by definition), each poll
// loop bounded.
#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kChains = 16;
constexpr unsigned kPollLimit = 1u << 22;

__device__ unsigned long long g_cycles[64];
__device__ double g_sink_d[1 << 16];
__device__ float g_sink_f[1 << 16];
__device__ unsigned g_sink_u[1 << 16];
__device__ int g_err;

// throughput: every thread kChains independent FMA chains, n steps
__global__ void dfma_rate(int n, double c, int lanes, int slot) {
  const int lane = threadIdx.x & 31;
  __syncthreads();
  const long long t0 = clock64();
  if (lane < lanes) {
    double y[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) y[k] = 1.0 + k + threadIdx.x;
    for (int i = 0; i < n; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) y[k] = fma(y[k], c, 0.25);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += y[k];
    g_sink_d[(blockIdx.x * blockDim.x + threadIdx.x) & 0xffff] = s;
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0 && blockIdx.x == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

__global__ void ffma_rate(int n, float c, int slot) {
  __syncthreads();
  const long long t0 = clock64();
  float y[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) y[k] = 1.0f + k + threadIdx.x;
  for (int i = 0; i < n; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) y[k] = fmaf(y[k], c, 0.25f);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += y[k];
  g_sink_f[(blockIdx.x * blockDim.x + threadIdx.x) & 0xffff] = s;
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0 && blockIdx.x == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

__global__ void imad_rate(int n, unsigned c, int slot) {
  __syncthreads();
  const long long t0 = clock64();
  unsigned y[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) y[k] = 1u + k + threadIdx.x;
  for (int i = 0; i < n; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) y[k] = y[k] * c + 7u;
  }
  unsigned s = 0u;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += y[k];
  g_sink_u[(blockIdx.x * blockDim.x + threadIdx.x) & 0xffff] = s;
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0 && blockIdx.x == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

// latency: one thread, one dependent chain
__global__ void dfma_latency(int n, double c, int slot) {
  if (threadIdx.x != 0) return;
  double y = 2.0;
  const long long t0 = clock64();
  for (int i = 0; i < n; ++i) y = fma(y, c, 0.25);
  const long long t1 = clock64();
  g_sink_d[0] = y;
  g_cycles[slot] = (unsigned long long)(t1 - t0);
}

// a double reciprocal square root fed by one multiply-add, dependent chain
__global__ void rsqrt_latency(int n, double c, int slot) {
  if (threadIdx.x != 0) return;
  double y = 2.0;
  const long long t0 = clock64();
  for (int i = 0; i < n; ++i) y = rsqrt(fma(y, c, 1.5));
  const long long t1 = clock64();
  g_sink_d[1] = y;
  g_cycles[slot] = (unsigned long long)(t1 - t0);
}

__global__ void barrier_cost(int n, int slot) {
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < n; ++i) __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned map_rank(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ unsigned ld_acquire(unsigned a) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned a, unsigned v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__global__ void __cluster_dims__(8, 1, 1) cluster_barrier_cost(int n, int slot) {
  cluster_barrier();
  const long long t0 = clock64();
  for (int i = 0; i < n; ++i) cluster_barrier();
  const long long t1 = clock64();
  if (threadIdx.x == 0 && cluster_rank() == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

// a flag in distributed shared memory passed back and forth between the two
// CTAs of a cluster (release store into the peer, acquire polls of its own)
__global__ void __cluster_dims__(2, 1, 1) dsmem_pingpong(int n, int slot) {
  __shared__ unsigned flag;
  if (threadIdx.x == 0) flag = 0u;
  cluster_barrier();
  const unsigned r = cluster_rank();
  const unsigned mine = map_rank(&flag, r), peer = map_rank(&flag, r ^ 1u);
  const long long t0 = clock64();
  if (threadIdx.x == 0) {
    for (unsigned i = 1; i <= (unsigned)n; ++i) {
      if (r == 0) st_release(peer, i);
      unsigned it = 0;
      while (ld_acquire(mine) != i && ++it < kPollLimit) {
      }
      if (it >= kPollLimit) {
        atomicExch(&g_err, 1);
        break;
      }
      if (r == 1) st_release(peer, i);
    }
  }
  const long long t1 = clock64();
  cluster_barrier();
  if (threadIdx.x == 0 && r == 0) g_cycles[slot] = (unsigned long long)(t1 - t0);
}

}  // namespace

int main() {
  int dev = 0, n_sm = 0, clk_khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const int n = 1024, nr = 256;
  for (int rep = 0; rep < 2; ++rep) {   // the first pass warms up, the second is kept
    dfma_rate<<<n_sm, 1024>>>(nr, 0.999, 32, 0);
    dfma_rate<<<n_sm, 1024>>>(nr, 0.999, 1, 1);
    ffma_rate<<<n_sm, 1024>>>(nr, 0.999f, 2);
    imad_rate<<<n_sm, 1024>>>(nr, 3u, 3);
    dfma_latency<<<1, 32>>>(n, 0.999, 4);
    rsqrt_latency<<<1, 32>>>(n, 0.999, 5);
    barrier_cost<<<1, 1024>>>(n, 6);
    barrier_cost<<<1, 256>>>(n, 7);
    cluster_barrier_cost<<<8, 256>>>(n, 8);
    dsmem_pingpong<<<2, 32>>>(n, 9);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      printf("{\"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
      return 1;
    }
  }
  // the same FP64 rate kernel timed by the wall clock (CUDA events), all SMs:
  // DFMA lanes per second, independent of what clock64() counts
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int nr_long = 4096;
  dfma_rate<<<n_sm, 1024>>>(nr_long, 0.999, 32, 10);
  cudaEventRecord(e0);
  dfma_rate<<<n_sm, 1024>>>(nr_long, 0.999, 32, 10);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const double dfma_per_s = (double)n_sm * 1024.0 * nr_long * kChains / (ms * 1e-3);
  unsigned long long c[64];
  int err = 0;
  cudaMemcpyFromSymbol(c, g_cycles, sizeof(c));
  cudaMemcpyFromSymbol(&err, g_err, sizeof(int));
  // warp instructions per SM in the rate kernels: 32 warps x nr x kChains
  const double winst = 32.0 * nr * kChains;
  const double ghz = clk_khz * 1e-6;
  auto lanes_per_clk = [&](unsigned long long cyc) { return winst * 32.0 / (double)cyc; };
  printf("{\"sm_count\": %d, \"sm_clock_ghz_nominal\": %.3f,\n", n_sm, ghz);
  printf(" \"dfma_lanes_per_clk_per_sm\": %.3f, \"dfma_cycles_per_warp_instr_per_sm\": %.2f,\n",
         lanes_per_clk(c[0]), c[0] / winst);
  printf(" \"dfma_one_lane_cycles_per_warp_instr_per_sm\": %.2f,\n", c[1] / winst);
  printf(" \"fp64_peak_gflops_at_nominal_clock\": %.1f,\n",
         lanes_per_clk(c[0]) * 2.0 * n_sm * ghz);
  printf(" \"ffma_lanes_per_clk_per_sm\": %.2f, \"imad_lanes_per_clk_per_sm\": %.2f,\n",
         lanes_per_clk(c[2]), lanes_per_clk(c[3]));
  printf(" \"dfma_dependent_latency_cycles\": %.1f, \"rsqrt_f64_plus_dfma_latency_cycles\": %.1f,\n",
         c[4] / (double)n, c[5] / (double)n);
  printf(" \"syncthreads_1024_cycles\": %.1f, \"syncthreads_256_cycles\": %.1f,\n", c[6] / (double)n,
         c[7] / (double)n);
  printf(" \"cluster8_barrier_cycles\": %.1f, \"dsmem_flag_round_trip_cycles\": %.1f,\n",
         c[8] / (double)n, c[9] / (double)n);
  printf(" \"dfma_per_s_events\": %.4g, \"dfma_lanes_per_clk_per_sm_events_at_nominal\": %.3f,\n",
         dfma_per_s, dfma_per_s / (n_sm * ghz * 1e9));
  printf(" \"dfma_cycles_long_run_per_warp_instr_per_sm\": %.2f,\n",
         c[10] / (32.0 * nr_long * kChains));
  printf(" \"poll_limit_hit\": %d}\n", err);
  return err ? 2 : 0;
}

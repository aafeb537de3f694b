// Self-test of the bounded device waits: the timeout path of tc::mbar_wait,
// run on purpose on an mbarrier that nothing arrives at (no fault, no hang).
#include "../../include/erx.h"
#include "erx_internal.cuh"
#include "tc_util.cuh"

namespace erx {
namespace {

__global__ void selftest_wait_kernel(uint32_t limit, unsigned long long* __restrict__ status) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);   // one arrival expected; none will come
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) *status = tc::mbar_wait(&mbar, 0u, limit) ? 1ull : 2ull;
}

}  // namespace
}  // namespace erx

using namespace erx;

extern "C" erx_status erx_selftest_bounded_wait(uint32_t limit, void* cuda_stream) {
  if (limit < 1 || limit > (1u << 20)) return ERX_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ENOMEM;
  }
  unsigned long long h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), st);
  if (e == cudaSuccess) {
    selftest_wait_kernel<<<1, 32, 0, st>>>(limit, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  return h == 2ull ? ERX_ETIMEOUT : h == 1ull ? ERX_OK : ERX_ECUDA;
}
